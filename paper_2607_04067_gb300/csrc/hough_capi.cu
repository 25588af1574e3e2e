// C ABI of libhough.so: argument checks, launch planning, workspace layout, CUDA-graph
// replay of the batched path, status words. See include/hough.h for the contract.
#include <cmath>
#include <cstring>
#include <algorithm>
#include <list>
#include <map>
#include <mutex>

#include "hough_internal.h"

namespace hgpu {

static thread_local int g_last_cuda = 0;
static thread_local cudaEvent_t g_ev_begin = nullptr, g_ev_end = nullptr;

static int cuda_fail(cudaError_t e) {
  g_last_cuda = (int)e;
  return HOUGH_ECUDA;
}

// Lets other files of the library report a CUDA error through hough_last_cuda_error.
void note_cuda_error(cudaError_t e) { g_last_cuda = (int)e; }

// th_j = (j + 1/2) pi / N_theta; c_j = round(2^14 cos th_j) (half away from zero).
void host_trig(int n_theta, TrigTable* t) {
  std::memset(t, 0, sizeof(*t));
  const double pi = 3.14159265358979323846;
  for (int j = 0; j < n_theta; ++j) {
    const double th = (j + 0.5) * pi / n_theta;
    t->c[j] = (int16_t)std::llround(16384.0 * std::cos(th));
    t->s[j] = (int16_t)std::llround(16384.0 * std::sin(th));
  }
}

// M = ceil(2^64 N_rho / 2H), split into 32-bit halves (M < 2^44 for N_rho <= 1024).
BinMagic host_magic(int n_rho) {
  const unsigned __int128 two_h = (unsigned __int128)(2 * kH);
  const unsigned __int128 num = ((unsigned __int128)1 << 64) * (unsigned __int128)n_rho;
  const unsigned __int128 M = (num + two_h - 1) / two_h;
  BinMagic m;
  m.lo = (uint32_t)(M & 0xffffffffu);
  m.hi = (uint32_t)(M >> 32);
  return m;
}

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

WsLayout ws_layout(const Plan& pl, long long n_events) {
  WsLayout w{};
  size_t o = 0;
  w.queue = o;
  o = align256(o + 64);
  const long long T = pl.tiles;
  w.tickets = o;
  if (T > 1) o = align256(o + 4 * (size_t)n_events);
  w.tile_cnt = o;  // per tile: record count and low-segment count
  if (T > 1) o = align256(o + 8 * (size_t)(n_events * T));
  w.tile_cs = o;
  if (T > 1) o = align256(o + 8 * (size_t)(n_events * T));
  w.tile_peaks = o;
  if (T > 1) o = align256(o + sizeof(hough_peak) * (size_t)(n_events * T) * (size_t)pl.max_peaks);
  const bool it_tiled = T > 1 && pl.peak_mode == HOUGH_PEAK_ITERATIVE;
  w.n_spill = it_tiled ? (int)std::min<long long>(std::max<long long>(n_events, 1), kSpillSlots) : 0;
  w.tile_max = o;
  if (it_tiled) o = align256(o + 4 * (size_t)(n_events * T));
  w.defer_list = o;
  if (it_tiled) o = align256(o + 4 * (size_t)(n_events > 0 ? n_events : 1));
  w.spill = o;
  if (it_tiled) o = align256(o + 4 * (size_t)w.n_spill * (size_t)pl.n_theta * (size_t)pl.n_rho);
  w.order = o;
  o = align256(o + 4 * (size_t)(n_events > 0 ? n_events : 1));
  w.total = o;
  return w;
}

void bind_workspace(const Plan& pl, const WsLayout& wl, char* ws, FusedIO& io) {
  const bool tiled = pl.tiles > 1, it_tiled = tiled && pl.peak_mode == HOUGH_PEAK_ITERATIVE;
  io.queue = (unsigned long long*)(ws + wl.queue);
  io.defer_count = (unsigned*)(ws + wl.queue + 8);  // reset with the queue counter by the validation kernel
  io.tickets = tiled ? (int*)(ws + wl.tickets) : nullptr;
  io.tile_cnt = tiled ? (int*)(ws + wl.tile_cnt) : nullptr;
  io.tile_cs = tiled ? (unsigned long long*)(ws + wl.tile_cs) : nullptr;
  io.tile_peaks = tiled ? (hough_peak*)(ws + wl.tile_peaks) : nullptr;
  io.tile_max = it_tiled ? (int*)(ws + wl.tile_max) : nullptr;
  io.defer_list = it_tiled ? (int*)(ws + wl.defer_list) : nullptr;
  io.spill = it_tiled ? (int*)(ws + wl.spill) : nullptr;
  io.n_spill = it_tiled ? wl.n_spill : 0;
}

static constexpr int kSmemBudget = 227 * 1024 - 2048;  // dynamic bytes; static shared memory stays below 2 KB

static int round16(int x) { return (x + 15) & ~15; }

// Shared-memory layout for a shape; returns false if it does not fit.
static bool layout(Plan& pl) {
  const int wpad = pl.groups * 32;
  const int cell = pl.acc32 ? 4 : 2;
  // mirror-pair: groups / 2 word groups of 32 lanes (the last may be part idle) x rows_phys
  const int acc_bytes = pl.mp ? (pl.groups / 2) * 32 * pl.rows_phys * 4 : wpad * pl.nrho_pad * cell;
  const int sel_bytes = (2 * pl.n_theta + 64) * 4 + pl.n_theta * 16 + pl.n_theta * pl.nrb_g * 4;
  int o = 0;
  pl.off_acc = o;
  pl.region_bytes = round16(acc_bytes > sel_bytes ? acc_bytes : sel_bytes);
  o += pl.region_bytes;
  pl.off_halo = o;
  if (pl.tiles > 1) o += round16(2 * (pl.mp ? pl.rows_phys : pl.nrho_pad) * 4);
  pl.off_hits = o;
  o += round16(pl.hit_cap * 8);
  pl.off_idx = o;
  if (pl.mp) o += round16(pl.hit_cap * 2);
  pl.off_pbits = o;  // also the iterative finder's slice and column maxima
  const bool it_whole = pl.peak_mode == HOUGH_PEAK_ITERATIVE && pl.tiles == 1;
  {
    int iter_words = 0;
    if (it_whole) {
      // candidate keys, then 2 state bits a cell (also room for the walk's 1-bit bitmap), then
      // two lists of undecided candidates (16-bit indices)
      const int cand_words = pl.iter_cap + (((pl.n_theta * pl.n_rho + 15) / 16 + 31) & ~31) + pl.iter_act;
      iter_words = iter_scratch_words(pl.n_theta, pl.n_rho, kIterSliceRows);
      if (pl.iter_cap > 0 && cand_words > iter_words) iter_words = cand_words;
    }
    o += round16((wpad * pl.nrb > iter_words ? wpad * pl.nrb : iter_words) * 4);
  }
  pl.off_cnt = o;  // record keys of the local-maximum scan or of a tile's candidates
  if (!it_whole) o += round16(wpad * pl.key_groups * 4);
  pl.off_unres = o;
  o += round16((pl.hit_cap + 1024) / 32 * 4);
  pl.off_trig = o;
  o += round16(2 * pl.n_theta * 2);
  pl.smem_bytes = o;
  if (o > kSmemBudget) return false;
  if (pl.peak_mode == HOUGH_PEAK_ITERATIVE && pl.tiles > 1) {
    // the merging CTA's candidates (a key and a state byte each, after the column starts) in
    // [off_acc, off_unres); the deferred kernel's finder (scratch, then a bitmap of every cell)
    // below the trig table
    const int free_bytes = pl.off_unres - pl.off_acc - 4 * ((pl.n_theta + 4) & ~3);
    pl.merge_cap = std::min(65520, free_bytes / 5) & ~15;  // key and state a candidate (16-bit indices)
    const int avail = pl.off_trig / 4, gone = (pl.n_theta * pl.n_rho + 31) / 32;
    int sh = kIterSliceRows;
    while (sh < pl.n_rho && iter_scratch_words(pl.n_theta, pl.n_rho, sh) + gone > avail) sh *= 2;
    const int sw = iter_scratch_words(pl.n_theta, pl.n_rho, sh);
    if (sw + gone > avail || pl.merge_cap < 64) return false;
    int cap = 16384;
    while (cap > 0 && (cap > sw ? cap : sw) + gone > avail) cap = cap > 1024 ? cap / 2 : 0;
    pl.def_sh = sh;
    pl.def_cap = cap;
  }
  return true;
}

static int check_params(const hough_params* p) {
  if (!p) return HOUGH_EINVAL;
  if (p->n_theta < 4 || p->n_theta > 1024 || p->n_rho < 4 || p->n_rho > 1024) return HOUGH_EPARAM;
  if (p->threshold < 1 || p->threshold > 32767) return HOUGH_EPARAM;
  if (p->keep_halfwidth < 0 || p->keep_halfwidth > 1024) return HOUGH_EPARAM;
  if (p->max_peaks < 1 || p->max_peaks > 65536) return HOUGH_EPARAM;
  if (p->theta_tiles < 0 || p->theta_tiles > 64 || p->theta_tiles > p->n_theta) return HOUGH_EPARAM;
  if (p->events_per_cta < 0 || p->events_per_cta > 1024) return HOUGH_EPARAM;
  if (p->block < 0 || p->block > 1024 || (p->block % 32) != 0) return HOUGH_EPARAM;
  if (p->peak_mode != HOUGH_PEAK_LOCAL_MAX && p->peak_mode != HOUGH_PEAK_ITERATIVE) return HOUGH_EPARAM;
  if (p->peak_mode == HOUGH_PEAK_ITERATIVE &&
      (p->rel_den < 1 || p->rel_num < 0 || p->rel_num > p->rel_den || p->nms_radius < 0 || p->nms_radius > 64 ||
       2 * p->nms_radius >= p->n_theta))
    return HOUGH_EPARAM;
  return HOUGH_OK;
}

// Constants of the mirror-pair vote's float row estimate k_f + 1 + 2^b + e (k_f = u A + v B +
// N_rho/2, 2^b > N_rho + 1, F = 23 - b fraction bits). Error bound of the estimate, in bins:
// A = fl(c fl(N_rho/2H)) is within 2^-23 (1 + 2^-24) of c N_rho/2H relative, and |u c| N_rho/2H
// <= (N_rho + 1)/2 for hits of the fast path (u^2 + v^2 <= lsq), so each product is off by
// at most (N_rho + 1) 2^-24 (1 + 2^-23); each of the two fused multiply-adds rounds a value
// in [2^b, 2^(b+1)) by at most 2^-(F+1). e (in units of 2^-F) is at least that bound and the
// ambiguous window [0, 2e) a power of two wide.
static void mp_consts(Plan& pl, int n_rho) {
  int b = 0;
  while ((1 << b) < n_rho + 2) ++b;
  const int F = 23 - b;
  pl.rows_phys = n_rho + 2;
  pl.mp_F = F;
  pl.mp_rmask = (1 << b) - 1;
  const double E = (n_rho + 1) * std::ldexp(1.0, F - 23) * (1.0 + std::ldexp(1.0, -20)) + 1.0;
  const int e_min = (int)std::ceil(E);
  int W = 2;
  while (W < 2 * e_min) W <<= 1;
  pl.mp_amask = ((1 << F) - 1) & ~(W - 1);
  pl.mp_k7 = (int)((uint32_t)((127 + b) << b) << 7);
  pl.mp_c0 = (float)(0.5 * n_rho + 1.0 + (double)(1 << b) + std::ldexp((double)(W / 2), -F));
  const double L = (double)kH * (1.0 + 1.0 / n_rho) / 16385.0;
  pl.mp_lsq = (long long)std::floor(L * L);
}

// Launch shape for parameters p; acc32 < 0 lets the planner choose the cell width.
int make_plan(const hough_params* p, Plan& pl, int acc32 = -1) {
  int rc = check_params(p);
  if (rc) return rc;
  std::memset(&pl, 0, sizeof(pl));
  pl.n_theta = p->n_theta;
  pl.n_rho = p->n_rho;
  pl.threshold = p->threshold;
  pl.keep_hw = p->keep_halfwidth;
  pl.max_peaks = p->max_peaks;
  pl.peak_mode = p->peak_mode;
  pl.rel_num = p->rel_num;
  pl.rel_den = p->rel_den;
  pl.nms_radius = p->nms_radius;
  pl.nrb = (p->n_rho + 31) / 32;
  pl.nrb_g = (p->n_rho + 2 + 31) / 32;
  pl.magic = host_magic(p->n_rho);
  pl.grab = p->events_per_cta > 0 ? p->events_per_cta : 1;
  {
    const double nr = p->n_rho, delta = nr * std::ldexp(1.0, -20);
    pl.fpbin = 1;
    pl.fp_scale = (float)(nr / (2.0 * (double)kH));
    pl.fp_c0 = (float)(0.5 * nr);
    pl.fp_khi = (float)(nr - 0.5);
    pl.fp_dlo = (float)(delta - 0.5);
    pl.fp_dhi = (float)(-delta - 0.5);
  }
  const int cell_choice = acc32 < 0 ? 0 : acc32;
  // Mirror pairs (columns j and N-1-j in one word) need an even N_theta and a table with
  // c[N-1-j] = -c[j], s[N-1-j] = s[j] (true for round-half-away-from-zero), int16 cells and
  // the float row estimate.
  bool sym = false;
  if (p->n_theta % 2 == 0 && !cell_choice && pl.fpbin) {
    TrigTable tt;
    host_trig(p->n_theta, &tt);
    sym = true;
    for (int j = 0; j < p->n_theta && sym; ++j)
      sym = tt.c[p->n_theta - 1 - j] == -tt.c[j] && tt.s[p->n_theta - 1 - j] == tt.s[j];
  }
  for (int T = (p->theta_tiles ? p->theta_tiles : 1); T <= (p->theta_tiles ? p->theta_tiles : 64); ++T) {
    // A mirror-pair tile owns WD = ceil(N/2 / T) words (columns [a, a + WD) and their mirrors;
    // the last tile fewer), in word groups of 32 lanes; other tiles W = ceil(N / T) columns.
    int W;
    if (sym) {
      const int NW = p->n_theta / 2, WD = (NW + T - 1) / T;
      if ((T - 1) * WD >= NW) continue;  // every tile must own at least one word
      W = 2 * WD;
      pl.groups = 2 * ((WD + 31) / 32);
    } else {
      W = (p->n_theta + T - 1) / T;
      if ((T - 1) * W >= p->n_theta) continue;  // every tile must own at least one column
      pl.groups = (W + 31) / 32;
    }
    pl.tiles = T;
    pl.tile_w = W;
    pl.acc32 = cell_choice;
    pl.nrho_pad = pl.acc32 ? p->n_rho : ((p->n_rho + 1) & ~1);
    const int halo = T > 1 ? 32 : 0;
    if (p->block) {
      const int work = p->block - halo;
      if (work <= 0 || work % (pl.groups * 32)) {
        if (p->theta_tiles) return HOUGH_EPARAM;
        continue;  // this tile count cannot use the requested block; try the next
      }
      pl.split = work / (pl.groups * 32);
    } else {
      // as many warps as fit 1024 threads: with one CTA per SM (large accumulators) the
      // extra warps hide the latency of the vote chains, the scan and the selection
      int s = (1024 - halo) / (pl.groups * 32);
      if (s < 1) s = 1;
      pl.split = s;
    }
    pl.threads = pl.groups * 32 * pl.split + halo;
    if (pl.threads > 1024) {
      if (p->theta_tiles) return HOUGH_EPARAM;
      continue;
    }
    pl.mirror = sym ? 1 : 0;
    pl.mp = pl.mirror;
    if (pl.mp) mp_consts(pl, p->n_rho);
    // row ranges of the peak scan: the power of two that minimises the slowest warp's row
    // steps, each unit (30 columns x one range) paying two extra rows to prime its window and
    // about 16 rows' worth of setup (measured at 256 x 256, 1024 threads: 4 ranges scan in
    // 9.4 k cycles an event, 8 in 9.5 k, 16 in 10.3 k, 32 in 12.6 k)
    {
      const bool packed = !pl.mp && !pl.acc32 && (p->n_rho & 1) == 0;
      const int cols = pl.mp ? pl.tile_w / 2 : pl.tile_w;
      const int nblk = (cols + 29) / 30, nwarps = pl.threads / 32;
      const int rows = packed ? p->n_rho / 2 : p->n_rho;
      long best = -1;
      for (int Rs = 0; (1 << Rs) <= 64 && (rows >> Rs) >= 2; ++Rs) {
        const long R = 1L << Rs;
        const long cost = ((nblk * R + nwarps - 1) / nwarps) * ((rows + R - 1) / R + 18);
        if (best < 0 || cost < best) {
          best = cost;
          pl.scan_ranges = (int)R;
          pl.scan_shift = Rs;
        }
      }
    }
    // keys of the peak records: (column, group of bitmap words), at most 4096 per CTA
    {
      int kg = 1, ks = 0;
      while (kg < pl.nrb) {
        kg <<= 1;
        ++ks;
      }
      int gw = 1;
      while (pl.groups * 32 * kg > 4096) {
        kg >>= 1;
        --ks;
        gw <<= 1;
      }
      pl.key_groups = kg;
      pl.key_shift = ks;
      pl.key_words = gw;
    }
    // the most staged hits, then (iterative finder) the most candidate keys of its candidate form
    for (int cap = 4096; cap >= 512; cap >>= 1) {
      pl.hit_cap = cap;
      const int icap0 = pl.peak_mode == HOUGH_PEAK_ITERATIVE && T == 1 ? 8192 : 0;
      for (int icap = icap0; icap >= 0; icap = icap > 1024 ? icap / 2 : icap - 1024) {
        pl.iter_cap = icap;
        for (int act = icap > 0 ? 2048 : 0; act >= 0;
             act = act > 1024 ? act - 512 : act > 256 ? act / 2 : act - 256) {  // 2048, 1536, 1024, 512, 256, 0
          pl.iter_act = act;
          if (layout(pl)) return HOUGH_OK;
        }
      }
    }
    if (p->theta_tiles) return HOUGH_ESMEM;
  }
  return HOUGH_ESMEM;
}

// ---- CUDA graph cache of the batched path ----

struct GraphKey {
  const void *xy, *off, *npeaks, *peaks, *mask, *nkept, *checksum, *ws, *status;
  long long n_hits, n_events;
  size_t ws_bytes;
  hough_params p;
  cudaStream_t stream;
  cudaEvent_t ev_begin, ev_end;
  int device;
  bool operator==(const GraphKey& o) const { return std::memcmp(this, &o, sizeof(GraphKey)) == 0; }
};

struct GraphEntry {
  GraphKey key;
  cudaGraphExec_t exec;
};

static std::mutex g_graph_mu;
static std::list<GraphEntry> g_graphs;

}  // namespace hgpu

using namespace hgpu;

namespace {

cudaError_t timed_fused(const Plan& pl, const FusedIO& io, const TrigTable& trig, int grid, cudaStream_t st) {
  cudaError_t e;
  // External records become real event-record nodes when the stream is being captured.
  if (g_ev_begin && g_ev_end) {
    e = cudaEventRecordWithFlags(g_ev_begin, st, cudaEventRecordExternal);
    if (e != cudaSuccess) return e;
  }
  e = launch_fused(pl, io, trig, grid, st);
  if (e == cudaSuccess && g_ev_begin && g_ev_end) e = cudaEventRecordWithFlags(g_ev_end, st, cudaEventRecordExternal);
  return e;
}

struct Common {
  Plan pl;
  WsLayout wl;
  FusedIO io;
};

int prepare_fused(const int32_t* d_xy, int64_t n_hits, const int64_t* d_off, int64_t n_events, const hough_params* p,
                  int32_t* d_npeaks, hough_peak* d_peaks, uint8_t* d_mask, int32_t* d_nkept, uint64_t* d_checksum,
                  void* d_ws, size_t ws_bytes, int32_t* d_status, Common& cm) {
  if (!d_off || !d_ws || !d_status) return HOUGH_EINVAL;
  if (n_hits < 0 || n_events < 0) return HOUGH_EINVAL;
  if (n_events > 0 && (!d_npeaks || !d_peaks || !d_nkept)) return HOUGH_EINVAL;
  if (n_hits > 0 && (!d_xy || !d_mask)) return HOUGH_EINVAL;
  if (((uintptr_t)d_xy & 7) || ((uintptr_t)d_peaks & 7) || ((uintptr_t)d_ws & 255)) return HOUGH_EINVAL;
  int rc = make_plan(p, cm.pl);
  if (rc) return rc;
  if ((long long)n_events * cm.pl.tiles > 0x7fffffffLL) return HOUGH_EINVAL;
  cm.wl = ws_layout(cm.pl, n_events);
  if (ws_bytes < cm.wl.total) return HOUGH_EWORKSPACE;
  char* ws = (char*)d_ws;
  FusedIO& io = cm.io;
  std::memset(&io, 0, sizeof(io));
  io.xy = (const int2*)d_xy;
  io.n_hits = n_hits;
  io.off = (const long long*)d_off;
  io.n_events = n_events;
  io.npeaks = d_npeaks;
  io.peaks = d_peaks;
  io.mask = d_mask;
  io.nkept = d_nkept;
  io.checksum = (unsigned long long*)d_checksum;
  io.status = d_status;
  bind_workspace(cm.pl, cm.wl, ws, io);
  io.n_items = n_events * (long long)cm.pl.tiles;
  return HOUGH_OK;
}

}  // namespace

extern "C" {

int hough_map(const int32_t* d_xy, int64_t n_hits, const int64_t* d_off, int64_t n_events, int64_t* d_uq,
              int64_t* d_vq, int32_t* d_status, void* stream) {
  if (!d_off || !d_status || n_hits < 0 || n_events < 0) return HOUGH_EINVAL;
  if (n_hits > 0 && (!d_xy || !d_uq || !d_vq)) return HOUGH_EINVAL;
  if ((uintptr_t)d_xy & 7) return HOUGH_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = launch_prep((const long long*)d_off, n_events, n_hits, d_status, nullptr, nullptr, nullptr, st);
  if (e != cudaSuccess) return cuda_fail(e);
  if (n_hits == 0) return HOUGH_OK;
  e = launch_map((const int2*)d_xy, n_hits, (long long*)d_uq, (long long*)d_vq, d_status, st);
  return e == cudaSuccess ? HOUGH_OK : cuda_fail(e);
}

int hough_vote(const int64_t* d_uq, const int64_t* d_vq, int64_t n_hits, const int64_t* d_off, int64_t n_events,
               const hough_params* p, int16_t* d_acc, int32_t* d_status, void* stream) {
  int rc = check_params(p);
  if (rc) return rc;
  if (!d_off || !d_status || n_hits < 0 || n_events < 0) return HOUGH_EINVAL;
  if (n_events > 0 && !d_acc) return HOUGH_EINVAL;
  if (n_hits > 0 && (!d_uq || !d_vq)) return HOUGH_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = launch_prep((const long long*)d_off, n_events, n_hits, d_status, nullptr, nullptr, nullptr, st);
  if (e != cudaSuccess) return cuda_fail(e);
  TrigTable trig;
  host_trig(p->n_theta, &trig);
  e = launch_vote((const long long*)d_uq, (const long long*)d_vq, (const long long*)d_off, n_events, *p, d_acc,
                  d_status, trig, st);
  return e == cudaSuccess ? HOUGH_OK : cuda_fail(e);
}

int hough_peaks(const int16_t* d_acc, int64_t n_events, const hough_params* p, int32_t* d_npeaks,
                hough_peak* d_peaks, int32_t* d_status, void* stream) {
  int rc = check_params(p);
  if (rc) return rc;
  if (!d_status || n_events < 0) return HOUGH_EINVAL;
  if (n_events > 0 && (!d_acc || !d_npeaks || !d_peaks)) return HOUGH_EINVAL;
  cudaError_t e = launch_peaks(d_acc, n_events, *p, d_npeaks, d_peaks, d_status, (cudaStream_t)stream);
  return e == cudaSuccess ? HOUGH_OK : cuda_fail(e);
}

int hough_select(const int64_t* d_uq, const int64_t* d_vq, int64_t n_hits, const int64_t* d_off, int64_t n_events,
                 const hough_params* p, const int32_t* d_npeaks, const hough_peak* d_peaks, uint8_t* d_mask,
                 int32_t* d_nkept, int32_t* d_status, void* stream) {
  int rc = check_params(p);
  if (rc) return rc;
  if (!d_off || !d_status || n_hits < 0 || n_events < 0) return HOUGH_EINVAL;
  if (n_events > 0 && (!d_npeaks || !d_peaks || !d_nkept)) return HOUGH_EINVAL;
  if (n_hits > 0 && (!d_uq || !d_vq || !d_mask)) return HOUGH_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = launch_prep((const long long*)d_off, n_events, n_hits, d_status, nullptr, nullptr, nullptr, st);
  if (e != cudaSuccess) return cuda_fail(e);
  TrigTable trig;
  host_trig(p->n_theta, &trig);
  e = launch_select((const long long*)d_uq, (const long long*)d_vq, (const long long*)d_off, n_events, *p, d_npeaks,
                    d_peaks, d_mask, d_nkept, d_status, trig, st);
  return e == cudaSuccess ? HOUGH_OK : cuda_fail(e);
}

int hough_circles(const int32_t* d_npeaks, const hough_peak* d_peaks, int64_t n_events, const hough_params* p,
                  double b_tesla, float* d_circles, void* stream) {
  int rc = check_params(p);
  if (rc) return rc;
  if (n_events < 0) return HOUGH_EINVAL;
  if (n_events > 0 && (!d_npeaks || !d_peaks || !d_circles)) return HOUGH_EINVAL;
  if (((uintptr_t)d_peaks & 7) || ((uintptr_t)d_circles & 15)) return HOUGH_EINVAL;
  const cudaError_t e = launch_circles(d_npeaks, d_peaks, n_events, p->n_theta, p->n_rho, p->max_peaks, b_tesla,
                                       d_circles, (cudaStream_t)stream);
  return e == cudaSuccess ? HOUGH_OK : cuda_fail(e);
}

size_t hough_workspace_size(const hough_params* p, int64_t n_events) {
  Plan pl;
  if (make_plan(p, pl) != HOUGH_OK || n_events < 0) return 256;
  return ws_layout(pl, n_events).total;
}

int hough_resolve_params(hough_params* p) {
  Plan pl;
  int rc = make_plan(p, pl);
  if (rc) return rc;
  p->theta_tiles = pl.tiles;
  p->events_per_cta = pl.grab;
  p->block = pl.threads;
  return HOUGH_OK;
}

int hough_run(const int32_t* d_xy, int64_t n_hits, const int64_t* d_off, int64_t n_events, const hough_params* p,
              int32_t* d_npeaks, hough_peak* d_peaks, uint8_t* d_mask, int32_t* d_nkept, uint64_t* d_checksum,
              void* d_ws, size_t ws_bytes, int32_t* d_status, void* stream) {
  Common cm;
  int rc = prepare_fused(d_xy, n_hits, d_off, n_events, p, d_npeaks, d_peaks, d_mask, d_nkept, d_checksum, d_ws,
                         ws_bytes, d_status, cm);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = launch_prep(cm.io.off, n_events, n_hits, d_status, cm.io.queue, cm.io.tickets, nullptr, st);
  if (e != cudaSuccess) return cuda_fail(e);
  if (cm.io.n_items == 0) return HOUGH_OK;
  TrigTable trig;
  host_trig(p->n_theta, &trig);
  cm.io.persistent = 0;
  e = timed_fused(cm.pl, cm.io, trig, (int)cm.io.n_items, st);
  return e == cudaSuccess ? HOUGH_OK : cuda_fail(e);
}

static int batched_grid(const Common& cm) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return -1;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return -1;
  const int per_sm = fused_max_ctas_per_sm(cm.pl);
  if (per_sm < 1) return -1;
  long long grid = (long long)sms * per_sm;
  if (grid > cm.io.n_items) grid = cm.io.n_items;
  return (int)(grid > 0 ? grid : 1);
}

static int enqueue_batched(const Common& cm0, const hough_params* p, int64_t n_hits, int64_t n_events, void* d_ws,
                           int32_t* d_status, int grid, cudaStream_t st) {
  Common cm = cm0;
  int* order = (int*)((char*)d_ws + cm.wl.order);
  cudaError_t e = launch_prep(cm.io.off, n_events, n_hits, d_status, cm.io.queue, cm.io.tickets, order, st);
  if (e != cudaSuccess) return cuda_fail(e);
  if (cm.io.n_items == 0) return HOUGH_OK;
  TrigTable trig;
  host_trig(p->n_theta, &trig);
  cm.io.order = order;
  cm.io.persistent = 1;
  e = timed_fused(cm.pl, cm.io, trig, grid, st);
  return e == cudaSuccess ? HOUGH_OK : cuda_fail(e);
}

// ---- autotuner ----

namespace {

// Everything but the launch shape that the work depends on, so that a cached shape is reused
// only for the same kind of work (the peak finder included).
struct TuneKey {
  int n_theta, n_rho, threshold, keep_hw, max_peaks, peak_mode, rel_num, rel_den, nms_radius, device, sms,
      hits_bucket;
  bool operator<(const TuneKey& o) const { return std::memcmp(this, &o, sizeof(TuneKey)) < 0; }
};

// The launch shape the autotuner picks; the rest of the caller's parameters is left alone.
struct TuneShape {
  int theta_tiles, events_per_cta, block;
};

std::mutex g_tune_mu;
std::map<TuneKey, TuneShape> g_tune_cache;

struct TuneScratch {
  size_t npeaks, peaks, mask, nkept, ws, total;
};

TuneScratch tune_scratch(const hough_params* p, int64_t n_hits, int64_t n_events) {
  TuneScratch L{};
  size_t o = 0;
  auto take = [&](size_t b) {
    const size_t at = o;
    o = (o + (b ? b : 1) + 255) & ~(size_t)255;
    return at;
  };
  L.npeaks = take(4 * (size_t)n_events);
  L.peaks = take(sizeof(hough_peak) * (size_t)n_events * (size_t)p->max_peaks);
  L.mask = take((size_t)n_hits);
  L.nkept = take(4 * (size_t)n_events);
  size_t ws = 0;
  for (int T = 1; T <= 16; T *= 2) {
    hough_params q = *p;
    q.theta_tiles = T;
    q.block = 0;
    Plan pl;
    if (make_plan(&q, pl) == HOUGH_OK) ws = std::max(ws, ws_layout(pl, n_events).total);
  }
  L.ws = take(ws);
  L.total = o;
  return L;
}

}  // namespace

size_t hough_autotune_scratch_size(const hough_params* p, int64_t n_hits, int64_t n_events) {
  if (check_params(p) != HOUGH_OK || n_hits < 0 || n_events < 0) return 256;
  return tune_scratch(p, n_hits, n_events).total;
}

int hough_autotune(hough_params* p, const int32_t* d_xy, int64_t n_hits, const int64_t* d_off, int64_t n_events,
                   void* d_scratch, size_t scratch_bytes, int32_t* d_status, void* stream, float* best_ms) {
  int rc = check_params(p);
  if (rc) return rc;
  if (!d_off || !d_scratch || !d_status || n_events < 1 || n_hits < 0 || ((uintptr_t)d_scratch & 255))
    return HOUGH_EINVAL;
  const TuneScratch L = tune_scratch(p, n_hits, n_events);
  if (scratch_bytes < L.total) return HOUGH_EWORKSPACE;
  TuneKey key;
  std::memset(&key, 0, sizeof(key));
  key.n_theta = p->n_theta;
  key.n_rho = p->n_rho;
  key.threshold = p->threshold;
  key.keep_hw = p->keep_halfwidth;
  key.max_peaks = p->max_peaks;
  key.peak_mode = p->peak_mode;
  key.rel_num = p->peak_mode == HOUGH_PEAK_ITERATIVE ? p->rel_num : 0;
  key.rel_den = p->peak_mode == HOUGH_PEAK_ITERATIVE ? p->rel_den : 0;
  key.nms_radius = p->peak_mode == HOUGH_PEAK_ITERATIVE ? p->nms_radius : 0;
  cudaGetDevice(&key.device);
  cudaDeviceGetAttribute(&key.sms, cudaDevAttrMultiProcessorCount, key.device);
  {
    const double hpe = (double)n_hits / (double)n_events;  // hit density in octaves
    int b = 0;
    while (b < 20 && (double)(1 << (b + 1)) <= hpe) ++b;
    key.hits_bucket = b;
  }
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
      p->theta_tiles = it->second.theta_tiles;
      p->events_per_cta = it->second.events_per_cta;
      p->block = it->second.block;
      if (best_ms) *best_ms = -1.0f;
      return HOUGH_OK;
    }
  }
  char* s = (char*)d_scratch;
  cudaStream_t st = (cudaStream_t)stream;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return cuda_fail(cudaGetLastError());
  hough_params best = *p;
  float best_t = 1e30f;
  bool found = false;
  for (int T = 1; T <= 16; T *= 2) {
    for (int threads : {256, 512, 1024}) {
      for (int grab : {1, 2, 4}) {
        hough_params q = *p;
        q.theta_tiles = T;
        q.events_per_cta = grab;
        Plan probe;
        q.block = 0;
        if (make_plan(&q, probe) != HOUGH_OK) continue;
        const int halo = T > 1 ? 32 : 0;
        const int lanes = probe.groups * 32;
        if (threads - halo <= 0 || (threads - halo) % lanes) {
          if (threads != 1024) continue;
          q.block = probe.threads;  // the widest block this tiling allows
        } else {
          q.block = threads;
        }
        Common cm;
        if (prepare_fused(d_xy, n_hits, d_off, n_events, &q, (int32_t*)(s + L.npeaks), (hough_peak*)(s + L.peaks),
                          (uint8_t*)(s + L.mask), (int32_t*)(s + L.nkept), nullptr, s + L.ws,
                          scratch_bytes - L.ws, d_status, cm) != HOUGH_OK)
          continue;
        const int grid = batched_grid(cm);
        if (grid < 1) continue;
        if (enqueue_batched(cm, &q, n_hits, n_events, s + L.ws, d_status, grid, st) != HOUGH_OK) continue;
        cudaEventRecord(e0, st);
        for (int r = 0; r < 2; ++r) enqueue_batched(cm, &q, n_hits, n_events, s + L.ws, d_status, grid, st);
        cudaEventRecord(e1, st);
        if (cudaEventSynchronize(e1) != cudaSuccess) continue;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        ms *= 0.5f;
        if (ms < best_t) {
          best_t = ms;
          best = q;
          found = true;
        }
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (!found) return HOUGH_ESMEM;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_cache[key] = TuneShape{best.theta_tiles, best.events_per_cta, best.block};
  }
  p->theta_tiles = best.theta_tiles;
  p->events_per_cta = best.events_per_cta;
  p->block = best.block;
  if (best_ms) *best_ms = best_t;
  return HOUGH_OK;
}

int hough_run_batched(const int32_t* d_xy, int64_t n_hits, const int64_t* d_off, int64_t n_events,
                      const hough_params* p, int32_t* d_npeaks, hough_peak* d_peaks, uint8_t* d_mask,
                      int32_t* d_nkept, uint64_t* d_checksum, void* d_ws, size_t ws_bytes, int32_t* d_status,
                      void* stream) {
  Common cm;
  int rc = prepare_fused(d_xy, n_hits, d_off, n_events, p, d_npeaks, d_peaks, d_mask, d_nkept, d_checksum, d_ws,
                         ws_bytes, d_status, cm);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  const int grid = batched_grid(cm);
  if (grid < 1) return HOUGH_ESMEM;
  if (st == nullptr) return enqueue_batched(cm, p, n_hits, n_events, d_ws, d_status, grid, st);  // legacy stream: no capture
  GraphKey key;
  std::memset(&key, 0, sizeof(key));
  key.xy = d_xy;
  key.off = d_off;
  key.npeaks = d_npeaks;
  key.peaks = d_peaks;
  key.mask = d_mask;
  key.nkept = d_nkept;
  key.checksum = d_checksum;
  key.ws = d_ws;
  key.status = d_status;
  key.n_hits = n_hits;
  key.n_events = n_events;
  key.ws_bytes = ws_bytes;
  key.p = *p;
  key.stream = st;
  key.ev_begin = g_ev_begin;
  key.ev_end = g_ev_end;
  cudaGetDevice(&key.device);
  std::lock_guard<std::mutex> lk(g_graph_mu);
  for (auto it = g_graphs.begin(); it != g_graphs.end(); ++it) {
    if (it->key == key) {
      g_graphs.splice(g_graphs.begin(), g_graphs, it);
      cudaError_t e = cudaGraphLaunch(it->exec, st);
      return e == cudaSuccess ? HOUGH_OK : cuda_fail(e);
    }
  }
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return cuda_fail(e);
  rc = enqueue_batched(cm, p, n_hits, n_events, d_ws, d_status, grid, st);
  e = cudaStreamEndCapture(st, &graph);
  if (rc) {
    if (graph) cudaGraphDestroy(graph);
    return rc;
  }
  if (e != cudaSuccess) return cuda_fail(e);
  cudaGraphExec_t exec = nullptr;
  e = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return cuda_fail(e);
  g_graphs.push_front(GraphEntry{key, exec});
  while (g_graphs.size() > 64) {
    cudaGraphExecDestroy(g_graphs.back().exec);
    g_graphs.pop_back();
  }
  e = cudaGraphLaunch(exec, st);
  return e == cudaSuccess ? HOUGH_OK : cuda_fail(e);
}

void hough_set_stage_events(void* begin, void* end) {
  g_ev_begin = (begin && end) ? (cudaEvent_t)begin : nullptr;
  g_ev_end = (begin && end) ? (cudaEvent_t)end : nullptr;
}

namespace {
constexpr int kHostChunks = 16;  // most event chunks of one hough_run_host call (measured: 4, 8, 16, 32)

struct HostLayout {
  size_t xy, off, npeaks, peaks, mask, nkept, peak_off, dense, ws, ws_bytes, total;
};

bool host_layout(const hough_params* p, int64_t n_hits, int64_t n_events, HostLayout& L) {
  Plan pl;
  if (make_plan(p, pl) != HOUGH_OK || n_hits < 0 || n_events < 0) return false;
  const size_t ne = (size_t)n_events, nh = (size_t)n_hits, mp = (size_t)p->max_peaks;
  size_t o = 0;
  auto take = [&](size_t bytes) {
    const size_t at = o;
    o = (o + (bytes ? bytes : 1) + 255) & ~(size_t)255;
    return at;
  };
  L.xy = take(8 * nh);
  L.off = take(8 * (ne + 1 + kHostChunks));  // per chunk its own rebased offsets
  L.npeaks = take(4 * ne);
  L.peaks = take(sizeof(hough_peak) * ne * mp);
  L.mask = take(nh);
  L.nkept = take(4 * ne);
  L.peak_off = take(8 * (ne + 1 + kHostChunks));
  L.dense = take(sizeof(hough_peak) * ne * mp);
  L.ws_bytes = ws_layout(pl, n_events).total;
  L.ws = take(L.ws_bytes);
  L.total = o;
  return true;
}
}  // namespace

size_t hough_host_buffer_size(const hough_params* p, int64_t n_hits, int64_t n_events) {
  HostLayout L;
  return host_layout(p, n_hits, n_events, L) ? L.total : 256;
}

// Timing events of one chunk, on the streams of their stages: copy-in [0, 1], kernels [2, 3],
// packing [3, 4], copy-out of counts, masks and offsets [5, 6], copy-out of the peaks [7, 8].
constexpr int kStageEvents = 9;

// Streams and events of the pipelined host path, per host thread and device.
struct HostPipe {
  int device = -1;
  cudaStream_t in = nullptr, out = nullptr, peaks = nullptr;
  cudaEvent_t ev[3 * kHostChunks] = {};
  bool ok = false;
  bool timing = false;  // per-stage timing of the calls on this thread (hough_set_host_timing)
  bool tev_ok = false;
  cudaEvent_t t_start = nullptr;
  cudaEvent_t tev[kStageEvents * kHostChunks] = {};
  float stage_ms[HOUGH_HOST_STAGES] = {};
  bool stage_valid = false;
};

static HostPipe& host_pipe_raw() {
  thread_local HostPipe hp;
  return hp;
}

static HostPipe& host_pipe() {
  HostPipe& hp = host_pipe_raw();
  int dev = 0;
  cudaGetDevice(&dev);
  if (!hp.ok || hp.device != dev) {
    hp.ok = cudaStreamCreateWithFlags(&hp.in, cudaStreamNonBlocking) == cudaSuccess &&
            cudaStreamCreateWithFlags(&hp.out, cudaStreamNonBlocking) == cudaSuccess &&
            cudaStreamCreateWithFlags(&hp.peaks, cudaStreamNonBlocking) == cudaSuccess;
    for (int i = 0; i < 3 * kHostChunks && hp.ok; ++i)
      hp.ok = cudaEventCreateWithFlags(&hp.ev[i], cudaEventDisableTiming) == cudaSuccess;
    hp.device = dev;
    hp.tev_ok = false;
  }
  if (hp.ok && hp.timing && !hp.tev_ok) {
    hp.tev_ok = cudaEventCreate(&hp.t_start) == cudaSuccess;
    for (int i = 0; i < kStageEvents * kHostChunks && hp.tev_ok; ++i) hp.tev_ok = cudaEventCreate(&hp.tev[i]) == cudaSuccess;
  }
  return hp;
}

// The batch is cut into up to kHostChunks event ranges that flow through four streams:
// copy-in (hits and offsets, rebased to the chunk), compute on `stream` (the batched path
// and the peak packing), copy-out (counts, mask, offsets) and, once a chunk's counts are on
// the host, a peak stream that copies exactly its stored peaks, so every transfer overlaps
// the kernels of other chunks.
int hough_run_host(const int32_t* h_xy, int64_t n_hits, const int64_t* h_off, int64_t n_events, const hough_params* p,
                   int32_t* h_npeaks, int64_t* h_peak_off, hough_peak* h_peaks, int64_t h_peaks_cap, uint8_t* h_mask,
                   int32_t* h_nkept, void* d_buf, size_t d_buf_bytes, int32_t* d_status, void* stream) {
  if (!h_off || !h_npeaks || !h_peak_off || !h_nkept || !d_buf || !d_status || n_hits < 0 || n_events < 0 ||
      h_peaks_cap < 0)
    return HOUGH_EINVAL;
  if (n_hits > 0 && (!h_xy || !h_mask)) return HOUGH_EINVAL;
  if (h_peaks_cap > 0 && !h_peaks) return HOUGH_EINVAL;
  if ((uintptr_t)d_buf & 255) return HOUGH_EINVAL;
  int rc = check_params(p);
  if (rc) return rc;
  HostLayout L;
  if (!host_layout(p, n_hits, n_events, L)) return HOUGH_EPARAM;
  if (d_buf_bytes < L.total) return HOUGH_EWORKSPACE;
  if (h_off[0] != 0 || h_off[n_events] != n_hits) return HOUGH_EINVAL;
  for (int64_t e = 0; e < n_events; ++e)
    if (h_off[e + 1] < h_off[e]) return HOUGH_EINVAL;
  HostPipe& hp = host_pipe();
  if (!hp.ok) return cuda_fail(cudaGetLastError());
  const bool timed = hp.timing && hp.tev_ok;
  hp.stage_valid = false;
  auto mark = [&](int c, int k, cudaStream_t s) {
    return timed ? cudaEventRecord(hp.tev[kStageEvents * c + k], s) : cudaSuccess;
  };
  char* b = (char*)d_buf;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t mp = (size_t)p->max_peaks;
  // chunk c: events [ce[c], ce[c + 1])
  const int K = (int)std::max<int64_t>(1, std::min<int64_t>(kHostChunks, n_events / 2048));
  int64_t ce[kHostChunks + 1];
  for (int c = 0; c <= K; ++c) ce[c] = n_events * c / K;
  cudaError_t e = cudaSuccess;
  int32_t* d_npk = (int32_t*)(b + L.npeaks);
  int32_t* d_nk = (int32_t*)(b + L.nkept);
  int64_t* d_off = (int64_t*)(b + L.off);
  int64_t* d_poff = (int64_t*)(b + L.peak_off);
  hough_peak* d_pk = (hough_peak*)(b + L.peaks);
  hough_peak* d_dense = (hough_peak*)(b + L.dense);
  uint8_t* d_mask = (uint8_t*)(b + L.mask);
  const int32_t* d_xy = (const int32_t*)(b + L.xy);
  // the compute stream's earlier work must not see half-written inputs: copy-in starts after it
  e = cudaEventRecord(hp.ev[0], st);
  if (e == cudaSuccess && timed) e = cudaEventRecord(hp.t_start, st);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(hp.in, hp.ev[0], 0);
  for (int c = 0; c < K && e == cudaSuccess; ++c) {
    const int64_t e0 = ce[c], n = ce[c + 1] - ce[c], a0 = h_off[e0], nh = h_off[ce[c + 1]] - a0;
    int64_t* roff = d_off + e0 + c;
    cudaEvent_t ev_in = hp.ev[3 * c], ev_comp = hp.ev[3 * c + 1], ev_out = hp.ev[3 * c + 2];
    e = mark(c, 0, hp.in);
    if (e == cudaSuccess) e = cudaMemcpyAsync(roff, h_off + e0, 8 * (size_t)(n + 1), cudaMemcpyHostToDevice, hp.in);
    if (e == cudaSuccess && nh)
      e = cudaMemcpyAsync((char*)d_xy + 8 * (size_t)a0, h_xy + 2 * a0, 8 * (size_t)nh, cudaMemcpyHostToDevice, hp.in);
    if (e == cudaSuccess) e = launch_rebase((long long*)roff, n + 1, a0, hp.in);
    if (e == cudaSuccess) e = mark(c, 1, hp.in);
    if (e == cudaSuccess) e = cudaEventRecord(ev_in, hp.in);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, ev_in, 0);
    if (e == cudaSuccess) e = mark(c, 2, st);
    if (e != cudaSuccess) break;
    rc = hough_run_batched(d_xy + 2 * a0, nh, roff, n, p, d_npk + e0, d_pk + e0 * mp, d_mask + a0, d_nk + e0,
                           nullptr, b + L.ws, L.ws_bytes, d_status, stream);
    if (rc) {  // nothing may still read or write the caller's host buffers after the return
      cudaStreamSynchronize(hp.in);
      cudaStreamSynchronize(hp.out);
      cudaStreamSynchronize(st);
      return rc;
    }
    e = mark(c, 3, st);
    if (e == cudaSuccess)
      e = launch_pack_peaks(d_npk + e0, d_pk + e0 * mp, n, p->max_peaks, (long long*)(d_poff + e0 + c),
                            d_dense + e0 * mp, st);
    if (e == cudaSuccess) e = mark(c, 4, st);
    if (e == cudaSuccess) e = cudaEventRecord(ev_comp, st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(hp.out, ev_comp, 0);
    if (e == cudaSuccess) e = mark(c, 5, hp.out);
    if (e == cudaSuccess && n) e = cudaMemcpyAsync(h_npeaks + e0, d_npk + e0, 4 * (size_t)n, cudaMemcpyDeviceToHost, hp.out);
    if (e == cudaSuccess && n) e = cudaMemcpyAsync(h_nkept + e0, d_nk + e0, 4 * (size_t)n, cudaMemcpyDeviceToHost, hp.out);
    if (e == cudaSuccess && nh) e = cudaMemcpyAsync(h_mask + a0, d_mask + a0, (size_t)nh, cudaMemcpyDeviceToHost, hp.out);
    if (e == cudaSuccess && n)
      e = cudaMemcpyAsync(h_peak_off + e0, d_poff + e0 + c, 8 * (size_t)n, cudaMemcpyDeviceToHost, hp.out);
    if (e == cudaSuccess) e = mark(c, 6, hp.out);
    if (e == cudaSuccess) e = cudaEventRecord(ev_out, hp.out);
  }
  // stored peaks, chunk by chunk, as each chunk's counts arrive
  int64_t base = 0;
  bool over = false;
  for (int c = 0; c < K && e == cudaSuccess; ++c) {
    const int64_t e0 = ce[c], n = ce[c + 1] - ce[c];
    e = cudaEventSynchronize(hp.ev[3 * c + 2]);
    if (e != cudaSuccess) break;
    int64_t tot = 0;
    for (int64_t i = e0; i < e0 + n; ++i) {
      h_peak_off[i] += base;
      tot += std::min<int64_t>(h_npeaks[i], (int64_t)mp);
    }
    if (base + tot > h_peaks_cap) over = true;
    // the chunk's packing finished before its counts were copied, which the host has seen
    e = mark(c, 7, hp.peaks);
    if (e == cudaSuccess && !over && tot > 0)
      e = cudaMemcpyAsync(h_peaks + base, d_dense + e0 * mp, sizeof(hough_peak) * (size_t)tot,
                          cudaMemcpyDeviceToHost, hp.peaks);
    if (e == cudaSuccess) e = mark(c, 8, hp.peaks);
    base += tot;
  }
  h_peak_off[n_events] = base;
  int32_t flags = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&flags, d_status, sizeof(int32_t), cudaMemcpyDeviceToHost, hp.out);
  // every stream is drained on every exit: no copy touches the caller's buffers afterwards
  const cudaError_t s1 = cudaStreamSynchronize(hp.in), s2 = cudaStreamSynchronize(hp.out);
  const cudaError_t s3 = cudaStreamSynchronize(hp.peaks), s4 = cudaStreamSynchronize(st);
  if (e == cudaSuccess) e = s1 != cudaSuccess ? s1 : s2 != cudaSuccess ? s2 : s3 != cudaSuccess ? s3 : s4;
  if (e != cudaSuccess) return cuda_fail(e);
  if (timed) {  // stage busy times summed over the chunks, and the span of the whole call
    float acc[HOUGH_HOST_STAGES] = {};
    float last = 0.f;
    bool ok = true;
    auto el = [&](cudaEvent_t a, cudaEvent_t z) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, a, z) != cudaSuccess) ok = false;
      return ms;
    };
    for (int c = 0; c < K && ok; ++c) {
      cudaEvent_t* t = hp.tev + kStageEvents * c;
      acc[HOUGH_HOST_STAGE_H2D] += el(t[0], t[1]);
      acc[HOUGH_HOST_STAGE_KERNELS] += el(t[2], t[3]);
      acc[HOUGH_HOST_STAGE_PACK] += el(t[3], t[4]);
      acc[HOUGH_HOST_STAGE_D2H] += el(t[5], t[6]);
      acc[HOUGH_HOST_STAGE_PEAKS_D2H] += el(t[7], t[8]);
      last = std::max(last, std::max(el(hp.t_start, t[6]), el(hp.t_start, t[8])));
    }
    acc[HOUGH_HOST_STAGE_SPAN] = last;
    cudaGetLastError();  // a failed elapsed-time query only invalidates the stage times
    if (ok) {
      std::memcpy(hp.stage_ms, acc, sizeof(acc));
      hp.stage_valid = true;
    }
  }
  if (over) return HOUGH_EWORKSPACE;
  return flags ? HOUGH_EDEVICE : HOUGH_OK;
}

void hough_set_host_timing(int32_t on) { host_pipe_raw().timing = on != 0; }

int hough_host_stage_ms(float* ms, int32_t n) {
  if (!ms || n < 0) return HOUGH_EINVAL;
  HostPipe& hp = host_pipe_raw();
  if (!hp.stage_valid) return HOUGH_EINVAL;
  for (int i = 0; i < n && i < HOUGH_HOST_STAGES; ++i) ms[i] = hp.stage_ms[i];
  return HOUGH_OK;
}

int hough_status(const int32_t* d_status, void* stream, int32_t* host_flags) {
  if (!d_status || !host_flags) return HOUGH_EINVAL;
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e);
  e = cudaMemcpy(host_flags, d_status, sizeof(int32_t), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e);
  return *host_flags ? HOUGH_EDEVICE : HOUGH_OK;
}

const char* hough_strerror(int code) {
  switch (code) {
    case HOUGH_OK: return "ok";
    case HOUGH_EINVAL: return "invalid argument (null pointer, negative count or misaligned buffer)";
    case HOUGH_EPARAM: return "parameters out of range";
    case HOUGH_ESMEM: return "shape does not fit shared memory";
    case HOUGH_ECUDA: return "CUDA runtime error";
    case HOUGH_EWORKSPACE: return "workspace too small";
    case HOUGH_ETIMEDOUT: return "bounded wait timed out";
    case HOUGH_EFULL: return "no free serving slot";
    case HOUGH_EDEVICE: return "device status flags set";
    case HOUGH_F_BAD_HIT: return "hit at r = 0 or beyond 2^24 um";
    case HOUGH_F_BAD_OFFSETS: return "event offsets invalid";
    case HOUGH_F_PEAK_OVERFLOW: return "more peaks than max_peaks";
    case HOUGH_F_EVENT_TOO_LARGE: return "event has more than HOUGH_MAX_EVENT_HITS hits";
    case HOUGH_F_TIMEOUT: return "micro-batch did not complete in time";
    case HOUGH_F_LAUNCH_FAILED: return "micro-batch could not be enqueued or failed on the device";
    default: return "unknown code";
  }
}

int hough_last_cuda_error(void) { return g_last_cuda; }

int hough_selftest_bin(int32_t n_rho, int64_t rho_lo, int64_t rho_hi, unsigned long long* d_mismatch,
                       void* stream) {
  if (!d_mismatch || n_rho < 4 || n_rho > 1024 || rho_hi < rho_lo) return HOUGH_EINVAL;
  cudaError_t e = launch_selftest_bin(n_rho, rho_lo, rho_hi, d_mismatch, (cudaStream_t)stream);
  return e == cudaSuccess ? HOUGH_OK : cuda_fail(e);
}

int hough_selftest_fpbin(int32_t n_theta, int32_t n_rho, uint64_t seed, int64_t n_samples, unsigned long long* d_out,
                         void* stream) {
  hough_params p{n_theta, n_rho, 1, 1, 1, 0, 0, 0, HOUGH_PEAK_LOCAL_MAX, 0, 1, 0};
  Plan pl;
  if (!d_out || n_samples < 0 || make_plan(&p, pl) != HOUGH_OK) return HOUGH_EINVAL;
  mp_consts(pl, n_rho);  // the mirror-pair estimate is checked whatever layout the plan chose
  TrigTable trig;
  host_trig(n_theta, &trig);
  cudaError_t e = launch_selftest_fpbin(pl, trig, seed, n_samples, d_out, (cudaStream_t)stream);
  return e == cudaSuccess ? HOUGH_OK : cuda_fail(e);
}

int hough_probe_smem_atomics(int32_t mode, int32_t ctas_per_sm, int32_t threads, int32_t smem_bytes, int32_t iters,
                             unsigned long long* d_sink, void* stream) {
  if (!d_sink || mode < 0 || mode > 4 || ctas_per_sm < 1 || threads < 32 || threads > 1024 || (threads % 32) ||
      smem_bytes < 4096 || smem_bytes > kSmemBudget || iters < 1)
    return HOUGH_EINVAL;
  cudaError_t e = launch_probe_atomics(mode, ctas_per_sm, threads, smem_bytes, iters, d_sink, (cudaStream_t)stream);
  return e == cudaSuccess ? HOUGH_OK : cuda_fail(e);
}

}  // extern "C"
