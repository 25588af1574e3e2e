// Stepwise kernels: the same path as the fused kernel, with every intermediate in HBM
// (u_q/v_q, the full int16 accumulator, the peak lists). They exist so that each step
// can be checked on its own against the CPU oracle; they favour plain code over speed.
#include <algorithm>
#include <climits>

#include "hough_internal.h"

namespace hgpu {
namespace {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// Conformal map, one thread per hit (Eq. 1-2). Bad hits get INT64_MIN.
__global__ void map_kernel(const int2* __restrict__ xy, long long n, long long* uq, long long* vq, int* status) {
  if (status[1] != 0) return;
  int bad = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int2 h = xy[i];
    long long u = 0, v = 0;
    if (map_hit(h.x, h.y, u, v)) {
      u = v = LLONG_MIN;
      bad = 1;
    }
    uq[i] = u;
    vq[i] = v;
  }
  bad = __syncthreads_or(bad);
  if (bad && threadIdx.x == 0) atomicOr(status, HOUGH_F_BAD_HIT);
}

// Voting, one CTA per (event, theta tile), one thread per theta column of the tile
// (Sec. 3: angle columns are independent, so a column owner needs no atomics).
__global__ void vote_kernel(const long long* __restrict__ uq, const long long* __restrict__ vq,
                            const long long* __restrict__ off, int NT, int NR, int T, int W, BinMagic m,
                            int16_t* __restrict__ acc, int* status, const TrigTable trig) {
  extern __shared__ int sacc[];  // [W][NR]
  if (status[1] != 0) return;
  const long long e = blockIdx.x / T;
  const int t = blockIdx.x % T;
  const int j0 = t * W, wt = min(W, NT - j0);
  const long long a = off[e], n = off[e + 1] - a;
  const bool big = n > HOUGH_MAX_EVENT_HITS;
  for (int i = threadIdx.x; i < wt * NR; i += blockDim.x) sacc[i] = 0;
  __syncthreads();
  const int c = threadIdx.x;
  if (!big && c < wt) {
    const long long cj = trig.c[j0 + c], sj = trig.s[j0 + c];
    int* col = sacc + c * NR;
    for (long long i = 0; i < n; ++i) {
      const long long u = uq[a + i], v = vq[a + i];
      if (u == LLONG_MIN) continue;
      col[rho_bin64(u * cj + v * sj + kH, m)] += 1;
    }
  }
  __syncthreads();
  int16_t* out = acc + (e * NT + j0) * (long long)NR;
  for (int i = threadIdx.x; i < wt * NR; i += blockDim.x) out[i] = (int16_t)sacc[i];
  if (big && threadIdx.x == 0) atomicOr(status, HOUGH_F_EVENT_TOO_LARGE);
}

// 3x3 rule for cell (j, k) of one event's accumulator A, read straight from HBM.
__device__ bool is_peak(const int16_t* A, int j, int k, int a, int NT, int NR) {
  for (int dj = -1; dj <= 1; ++dj) {
    for (int dk = -1; dk <= 1; ++dk) {
      if (dj == 0 && dk == 0) continue;
      int kk = k + dk, jj = j + dj;
      if (kk < 0 || kk >= NR) continue;
      if (jj < 0) {
        jj = NT - 1;
        kk = NR - 1 - kk;
      } else if (jj >= NT) {
        jj = 0;
        kk = NR - 1 - kk;
      }
      const int b = A[jj * NR + kk];
      const bool prec = (jj * NR + kk) < (j * NR + k);
      if (prec ? !(a > b) : !(a >= b)) return false;
    }
  }
  return true;
}

// Peaks of one event per CTA, cells visited in raster order, ordered compaction.
__global__ void peaks_kernel(const int16_t* __restrict__ acc, int NT, int NR, int thr, int maxp, int* npeaks,
                             hough_peak* peaks, int* status) {
  __shared__ int s_w[32];
  __shared__ int s_base;
  const long long e = blockIdx.x;
  const int16_t* A = acc + e * (long long)NT * NR;
  const int ncell = NT * NR, lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (threadIdx.x == 0) s_base = 0;
  __syncthreads();
  for (int c0 = 0; c0 < ncell; c0 += blockDim.x) {
    const int cidx = c0 + threadIdx.x;
    bool pk = false;
    int j = 0, k = 0, a = 0;
    if (cidx < ncell) {
      j = cidx / NR;
      k = cidx % NR;
      a = A[cidx];
      pk = a >= thr && is_peak(A, j, k, a, NT, NR);
    }
    const unsigned bal = __ballot_sync(kFull, pk);
    if (lane == 0) s_w[w] = __popc(bal);
    __syncthreads();
    int before = 0, tot = 0;
    for (int i = 0; i < nw; ++i) {
      if (i < w) before += s_w[i];
      tot += s_w[i];
    }
    const int pos = s_base + before + __popc(bal & lanemask_lt());
    if (pk && pos < maxp) {
      hough_peak q;
      q.theta_bin = (int16_t)j;
      q.rho_bin = (int16_t)k;
      q.votes = (int16_t)a;
      q.flags = 0;
      peaks[e * maxp + pos] = q;
    }
    __syncthreads();
    if (threadIdx.x == 0) s_base += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    npeaks[e] = s_base;
    if (s_base > maxp) atomicOr(status, HOUGH_F_PEAK_OVERFLOW);
  }
}

// Selection, one CTA per event, one thread per hit, every stored peak tried in turn.
__global__ void select_kernel(const long long* __restrict__ uq, const long long* __restrict__ vq,
                              const long long* __restrict__ off, int NT, int NR, int hw, int maxp, BinMagic m,
                              const int* npeaks, const hough_peak* __restrict__ peaks, uint8_t* mask, int* nkept,
                              int* status, const TrigTable trig) {
  __shared__ int s_kept;
  if (status[1] != 0) return;
  const long long e = blockIdx.x;
  const long long a = off[e], n = off[e + 1] - a;
  const bool big = n > HOUGH_MAX_EVENT_HITS;
  const int S = big ? 0 : min(npeaks[e], maxp);
  const hough_peak* pk = peaks + e * maxp;
  if (threadIdx.x == 0) s_kept = 0;
  __syncthreads();
  int kept = 0;
  for (long long i = threadIdx.x; i < n; i += blockDim.x) {
    const long long u = uq[a + i], v = vq[a + i];
    int keep = 0;
    if (u != LLONG_MIN) {
      for (int q = 0; q < S && !keep; ++q) {
        const hough_peak p = pk[q];
        if (p.theta_bin < 0 || p.theta_bin >= NT) continue;  // caller-supplied list: ignore foreign columns
        const int k = rho_bin64(u * trig.c[p.theta_bin] + v * trig.s[p.theta_bin] + kH, m);
        keep = abs(k - (int)p.rho_bin) <= hw;
      }
    }
    mask[a + i] = (uint8_t)keep;
    kept += keep;
  }
  for (int o = 16; o > 0; o >>= 1) kept += __shfl_down_sync(kFull, kept, o);
  if ((threadIdx.x & 31) == 0 && kept) atomicAdd(&s_kept, kept);
  __syncthreads();
  if (threadIdx.x == 0) nkept[e] = s_kept;
}

// Offsets of each event's stored peaks in a dense list (single CTA, sequential chunks).
__global__ void __launch_bounds__(1024) pack_offsets_kernel(const int* npeaks, long long ne, int maxp,
                                                            long long* peak_off) {
  __shared__ long long s_w[32];
  __shared__ long long s_carry;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (threadIdx.x == 0) s_carry = 0;
  __syncthreads();
  for (long long b = 0; b < ne; b += blockDim.x) {
    const long long e = b + threadIdx.x;
    const long long c = e < ne ? (long long)min(npeaks[e], maxp) : 0;
    long long x = c;
    for (int o = 1; o < 32; o <<= 1) {
      const long long y = __shfl_up_sync(kFull, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) s_w[w] = x;
    __syncthreads();
    long long before = s_carry;
    for (int i = 0; i < w; ++i) before += s_w[i];
    if (e < ne) peak_off[e] = before + x - c;
    __syncthreads();
    if (threadIdx.x == 0) {
      long long t = 0;
      for (int i = 0; i < nw; ++i) t += s_w[i];
      s_carry += t;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) peak_off[ne] = s_carry;
}

__global__ void pack_copy_kernel(const int* npeaks, const hough_peak* __restrict__ peaks, long long ne, int maxp,
                                 const long long* peak_off, hough_peak* dense) {
  for (long long e = blockIdx.x; e < ne; e += gridDim.x) {
    const int c = min(npeaks[e], maxp);
    const int2* src = reinterpret_cast<const int2*>(peaks + e * maxp);
    int2* dst = reinterpret_cast<int2*>(dense + peak_off[e]);
    for (int i = threadIdx.x; i < c; i += blockDim.x) dst[i] = src[i];
  }
}

// Exhaustive check of the device bin function: each thread walks a contiguous rho range
// and tracks the exact bin by integer bin boundaries (one division per boundary).
__global__ void selftest_bin_kernel(int NR, BinMagic m, long long lo, long long hi, unsigned long long* mism) {
  const long long total = hi - lo + 1;
  const long long nth = (long long)gridDim.x * blockDim.x;
  const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long per = (total + nth - 1) / nth;
  const long long r0 = lo + tid * per, r1 = min(hi + 1, r0 + per);
  unsigned long long bad = 0;
  if (r0 < r1) {
    const long long two_h = 2 * kH;
    auto exact = [&](long long t) -> long long {
      return t < 0 ? 0 : min((long long)NR - 1, (t * NR) / two_h);
    };
    long long ref = exact(r0 + kH);
    // smallest t with exact(t) > ref (only meaningful while ref < NR - 1 and t >= 0)
    auto next_edge = [&](long long k) -> long long { return ((k + 1) * two_h + NR - 1) / NR; };
    long long edge = (r0 + kH < 0) ? 0 : next_edge(ref);
    for (long long rho = r0; rho < r1; ++rho) {
      const long long t = rho + kH;
      if (t >= edge && ref < NR - 1) {
        ref = exact(t);
        edge = next_edge(ref);
      }
      bad += (rho_bin64(t, m) != ref);
    }
  }
  for (int o = 16; o > 0; o >>= 1) bad += __shfl_down_sync(kFull, bad, o);
  if ((threadIdx.x & 31) == 0 && bad) atomicAdd(mism, bad);
}

// Shared-memory atomic throughput: 16 register-held addresses per thread, red.shared.add
// issued back to back.
__global__ void probe_kernel(int mode, int words, int iters, unsigned long long* sink) {
  extern __shared__ uint32_t sm[];
  for (int i = threadIdx.x; i < words; i += blockDim.x) sm[i] = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int rows = words >> 5;
  uint32_t* p[16];
#pragma unroll
  for (int r = 0; r < 16; ++r) {
    int w;
    if (mode == 0) {
      w = ((warp * 16 + r) % rows) * 32 + lane;
    } else if (mode == 1) {
      unsigned long long z = (unsigned long long)(blockIdx.x * 1315423911u + threadIdx.x * 2654435761u + r * 97u);
      w = (int)(mix64(z) % (unsigned long long)words);
    } else if (mode == 2) {
      w = ((warp * 16 + r) % rows) * 32;
    } else if (mode == 3) {
      w = (warp % rows) * 32 + lane;  // each thread keeps adding to one word of its own bank
    } else {  // mode 4: each lane on its own bank, at pseudo-random rows (the vote's pattern)
      unsigned long long z = (unsigned long long)(blockIdx.x * 2654435761u + threadIdx.x * 40503u + r * 97u);
      w = (int)(mix64(z) % (unsigned long long)rows) * 32 + lane;
    }
    p[r] = sm + w;
  }
  const uint32_t inc = (mode == 1) ? (1u << ((lane & 1) << 4)) : 1u;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int r = 0; r < 16; ++r) red_add_shared(p[r], inc);
  }
  __syncthreads();
  if (threadIdx.x == 0) atomicAdd(sink, (unsigned long long)sm[blockIdx.x % words]);
}

// Circle of each stored peak (Eq. 2 at the bin centres), one thread per record.
__global__ void circles_kernel(const int* __restrict__ npeaks, const hough_peak* __restrict__ peaks,
                               long long n_events, int n_theta, int n_rho, int max_peaks, double b_tesla,
                               float4* __restrict__ out) {
  const long long total = n_events * (long long)max_peaks;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const long long e = i / max_peaks;
    const int q = (int)(i - e * max_peaks);
    if (q >= min(npeaks[e], max_peaks)) continue;
    const hough_peak pk = peaks[i];
    double sn, cs;
    sincospi(((double)pk.theta_bin + 0.5) / (double)n_theta, &sn, &cs);
    const double rho = (-1.0 + (2.0 * (double)pk.rho_bin + 1.0) / (double)n_rho) * 0.01;
    const double rc = 1.0 / fabs(rho);
    out[i] = make_float4((float)(cs / rho), (float)(sn / rho), (float)rc, (float)(0.3 * b_tesla * rc));
  }
}

// The iterative finder on an accumulator in HBM (read only): suppressed cells are kept in a
// shared-memory bitmap, one CTA per event.
struct GlobalCells {
  static constexpr bool kPairs = false;
  const int16_t* A;
  uint32_t* gone;
  int NR;
  __device__ int get(int j, int k) const {
    const int c = j * NR + k;
    return ((gone[c >> 5] >> (c & 31)) & 1u) ? 0 : (int)A[c];
  }
  __device__ void clear(int j, int k) {
    const int c = j * NR + k;
    atomicOr(&gone[c >> 5], 1u << (c & 31));
  }
};

__global__ void peaks_iterative_kernel(const int16_t* __restrict__ acc, int NT, int NR, int SH, int cap, int thr,
                                       int rel_num, int rel_den, int R, int maxp, int* npeaks, hough_peak* peaks,
                                       int* status) {
  extern __shared__ uint32_t sm[];
  __shared__ int s_sel[8];
  const long long e = blockIdx.x;
  // the finder's scratch, then the suppression bitmap (also the candidate walk's bitmap)
  const int sw = iter_scratch_words(NT, NR, SH);
  uint32_t* cm = sm;
  uint32_t* gone = sm + (sw > cap ? sw : cap);
  const int nwords = (NT * NR + 31) >> 5;
  for (int i = threadIdx.x; i < nwords; i += blockDim.x) gone[i] = 0u;
  __syncthreads();
  GlobalCells cells{acc + e * (long long)NT * NR, gone, NR};
  const int n =
      extract_iterative(cells, NT, NR, SH, thr, rel_num, rel_den, R, maxp, cm, cap, gone, 0, peaks + e * maxp, s_sel);
  if (threadIdx.x == 0) {
    npeaks[e] = n;
    if (n > maxp) atomicOr(status, HOUGH_F_PEAK_OVERFLOW);
  }
}

// Offsets of a chunk of a batch, made relative to the chunk's first hit.
__global__ void rebase_kernel(long long* off, long long n, long long a0) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    off[i] -= a0;
}

}  // namespace

cudaError_t launch_map(const int2* xy, long long n_hits, long long* uq, long long* vq, int* status, cudaStream_t st) {
  long long blocks = (n_hits + 255) / 256;
  if (blocks < 1) blocks = 1;
  if (blocks > 65535LL * 16) blocks = 65535LL * 16;
  map_kernel<<<(unsigned)blocks, 256, 0, st>>>(xy, n_hits, uq, vq, status);
  return cudaGetLastError();
}

cudaError_t launch_vote(const long long* uq, const long long* vq, const long long* off, long long n_events,
                        const hough_params& p, int16_t* acc, int* status, const TrigTable& trig, cudaStream_t st) {
  if (n_events == 0) return cudaSuccess;
  const int NT = p.n_theta, NR = p.n_rho;
  int T = 1;
  while ((long long)((NT + T - 1) / T) * NR * 4 > 160 * 1024) ++T;
  const int W = (NT + T - 1) / T;
  const int threads = ((W + 31) / 32) * 32;
  const int smem = W * NR * 4;
  cudaError_t err = cudaFuncSetAttribute((const void*)vote_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (err != cudaSuccess) return err;
  vote_kernel<<<(unsigned)(n_events * T), threads, smem, st>>>(uq, vq, off, NT, NR, T, W, host_magic(NR), acc, status,
                                                               trig);
  return cudaGetLastError();
}

cudaError_t launch_peaks(const int16_t* acc, long long n_events, const hough_params& p, int* npeaks,
                         hough_peak* peaks, int* status, cudaStream_t st) {
  if (n_events == 0) return cudaSuccess;
  if (p.peak_mode == HOUGH_PEAK_ITERATIVE) {
    // slices of 32 rows, or taller ones where the maxima and the suppression bitmap would not
    // fit in shared memory; then as many candidate keys for the candidate form as the rest holds
    const int nwords = (p.n_theta * p.n_rho + 31) / 32, budget = 200 * 1024 / 4;
    int SH = 32;
    while (iter_scratch_words(p.n_theta, p.n_rho, SH) + nwords > budget) SH *= 2;
    const int sw = iter_scratch_words(p.n_theta, p.n_rho, SH);
    int cap = 16384;
    while (cap > 0 && (cap > sw ? cap : sw) + nwords > budget) cap = cap > 1024 ? cap / 2 : 0;
    const int smem = ((cap > sw ? cap : sw) + nwords) * 4;
    cudaError_t err = cudaFuncSetAttribute((const void*)peaks_iterative_kernel,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (err != cudaSuccess) return err;
    peaks_iterative_kernel<<<(unsigned)n_events, 512, smem, st>>>(acc, p.n_theta, p.n_rho, SH, cap, p.threshold,
                                                                  p.rel_num, p.rel_den, p.nms_radius, p.max_peaks,
                                                                  npeaks, peaks, status);
    return cudaGetLastError();
  }
  peaks_kernel<<<(unsigned)n_events, 256, 0, st>>>(acc, p.n_theta, p.n_rho, p.threshold, p.max_peaks, npeaks, peaks,
                                                   status);
  return cudaGetLastError();
}

cudaError_t launch_select(const long long* uq, const long long* vq, const long long* off, long long n_events,
                          const hough_params& p, const int* npeaks, const hough_peak* peaks, uint8_t* mask,
                          int* nkept, int* status, const TrigTable& trig, cudaStream_t st) {
  if (n_events == 0) return cudaSuccess;
  select_kernel<<<(unsigned)n_events, 256, 0, st>>>(uq, vq, off, p.n_theta, p.n_rho, p.keep_halfwidth, p.max_peaks,
                                                    host_magic(p.n_rho), npeaks, peaks, mask, nkept, status, trig);
  return cudaGetLastError();
}

cudaError_t launch_circles(const int* npeaks, const hough_peak* peaks, long long n_events, int n_theta, int n_rho,
                           int max_peaks, double b_tesla, float* circles, cudaStream_t st) {
  const long long total = n_events * (long long)max_peaks;
  if (total == 0) return cudaSuccess;
  const long long blocks = min((total + 255) / 256, 152LL * 16);
  circles_kernel<<<(unsigned)blocks, 256, 0, st>>>(npeaks, peaks, n_events, n_theta, n_rho, max_peaks, b_tesla,
                                                   reinterpret_cast<float4*>(circles));
  return cudaGetLastError();
}

cudaError_t launch_rebase(long long* off, long long n, long long a0, cudaStream_t st) {
  if (n <= 0 || a0 == 0) return cudaSuccess;
  const long long blocks = std::min<long long>((n + 255) / 256, 152LL * 8);
  rebase_kernel<<<(unsigned)blocks, 256, 0, st>>>(off, n, a0);
  return cudaGetLastError();
}

cudaError_t launch_pack_peaks(const int* npeaks, const hough_peak* peaks, long long n_events, int max_peaks,
                              long long* peak_off, hough_peak* dense, cudaStream_t st) {
  pack_offsets_kernel<<<1, 1024, 0, st>>>(npeaks, n_events, max_peaks, peak_off);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || n_events == 0) return e;
  const long long grid = n_events < 152 * 16 ? n_events : 152 * 16;
  pack_copy_kernel<<<(unsigned)grid, 256, 0, st>>>(npeaks, peaks, n_events, max_peaks, peak_off, dense);
  return cudaGetLastError();
}

cudaError_t launch_selftest_bin(int n_rho, long long lo, long long hi, unsigned long long* mismatch, cudaStream_t st) {
  selftest_bin_kernel<<<152 * 8, 256, 0, st>>>(n_rho, host_magic(n_rho), lo, hi, mismatch);
  return cudaGetLastError();
}

cudaError_t launch_probe_atomics(int mode, int ctas_per_sm, int threads, int smem_bytes, int iters,
                                 unsigned long long* sink, cudaStream_t st) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaError_t err =
      cudaFuncSetAttribute((const void*)probe_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes);
  if (err != cudaSuccess) return err;
  probe_kernel<<<sms * ctas_per_sm, threads, smem_bytes, st>>>(mode, smem_bytes / 4, iters, sink);
  return cudaGetLastError();
}

}  // namespace hgpu
