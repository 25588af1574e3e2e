// Library-internal declarations shared by the kernel files and the C ABI layer.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "hough.h"
#include "hough_device.cuh"

namespace hgpu {

// Rows per slice of the iterative finder's slice maxima in the fused kernel.
constexpr int kIterSliceRows = 32;

// Launch shape and shared-memory layout of the fused kernel for one parameter set.
struct Plan {
  int n_theta, n_rho, threshold, keep_hw, max_peaks;
  int peak_mode, rel_num, rel_den, nms_radius;  // peak finder (0: 3x3 local maxima, 1: iterative)
  int iter_cap;   // iterative finder: candidate keys of its candidate form (0: one pass per peak only)
  int iter_act;   // iterative finder: entries of each of its two lists of undecided candidates
  int tiles;      // theta tiles per event
  int tile_w;     // columns per tile (last tile may be narrower)
  int groups;     // 32-column groups per tile
  int split;      // warps voting each column group (hit partitions)
  int threads;    // CTA size: groups * split * 32 (+ 32 halo lanes when tiles > 1)
  int acc32;      // 1: one int32 cell per shared word; 0: two int16 cells per word
  int nrho_pad;   // rows allocated per column
  int nrb;        // 32-bit bitmap words per column
  int nrb_g;      // bitmap words per column with one guard bit on each side
  int hit_cap;    // hits staged in shared memory per chunk
  int scan_ranges;  // row ranges of the peak scan (a power of two)
  int scan_shift;   // log2(scan_ranges)
  int key_groups;   // peak-record keys per column (a power of two)
  int key_shift;    // log2(key_groups)
  int key_words;    // bitmap words per key
  int grab;       // persistent queue: items per pop
  int mirror;     // 1: each vote lane owns column j and its mirror N_theta-1-j
  int fpbin;      // 1: fast-path bins from a float estimate, exact integer path when ambiguous
  int mp;         // 1: mirror-pair word layout (column j low half, N_theta-1-j high half, guard rows)
  int rows_phys;  // mirror-pair layout: physical rows per column (N_rho + 2)
  int mp_F, mp_rmask, mp_amask, mp_k7;  // float row estimate: fraction bits, row mask, ambiguity mask,
                                        // exponent bits of (y >> F) << 7
  float mp_c0;    // N_rho/2 + 1 + 2^b + W/2 2^-F
  long long mp_lsq;  // fast path when u^2 + v^2 <= mp_lsq (rho within half a bin of the range)
  float fp_scale, fp_c0, fp_khi, fp_dlo, fp_dhi;  // N_rho/2H, N_rho/2, N_rho-1/2, delta-1/2, -delta-1/2
  // iterative finder on theta tiles: candidate keys the merging CTA holds; slice height and
  // candidate keys of the deferred kernel's finder
  int merge_cap, def_sh, def_cap;
  // shared-memory layout in bytes
  int off_acc, region_bytes, off_halo, off_hits, off_idx, off_pbits, off_cnt, off_unres, off_trig, smem_bytes;
  BinMagic magic;
};

struct FusedIO {
  const int2* xy;
  long long n_hits;
  const long long* off;
  long long n_events;
  int* npeaks;
  hough_peak* peaks;
  uint8_t* mask;
  int* nkept;
  unsigned long long* checksum;  // nullable
  int* status;                   // [0] sticky flags, [1] per-call offsets flag
  unsigned long long* queue;     // persistent item counter
  const int* order;              // nullable: events in processing order
  int* tickets;                  // per event, tiles > 1
  int* tile_cnt;                 // [n_events * tiles]
  unsigned long long* tile_cs;   // [n_events * tiles]
  hough_peak* tile_peaks;        // [n_events * tiles * max_peaks]
  // iterative finder on theta tiles: each tile's maximum, the events deferred to the fallback
  // kernel (count, list) and its accumulators in HBM (n_spill of n_theta * n_rho int32 cells)
  int* tile_max;                 // [n_events * tiles]
  unsigned* defer_count;
  int* defer_list;               // [n_events]
  int* spill;
  int n_spill;
  long long n_items;
  int persistent;
};

// Workspace carve-up (byte offsets inside the caller's buffer).
struct WsLayout {
  size_t queue, tickets, tile_cnt, tile_cs, tile_peaks, tile_max, defer_list, spill, order, total;
  int n_spill;
};

// Accumulators in HBM for events the tiled iterative finder defers (at most this many at once).
constexpr int kSpillSlots = 8;

WsLayout ws_layout(const Plan& pl, long long n_events);
// Points the workspace fields of io into ws (laid out by wl) and clears the others.
void bind_workspace(const Plan& pl, const WsLayout& wl, char* ws, FusedIO& io);
void host_trig(int n_theta, TrigTable* t);
BinMagic host_magic(int n_rho);

cudaError_t launch_prep(const long long* off, long long n_events, long long n_hits, int* status,
                        unsigned long long* queue, int* tickets, int* order, cudaStream_t st);
cudaError_t launch_fused(const Plan& pl, const FusedIO& io, const TrigTable& trig, int grid, cudaStream_t st);
int fused_max_ctas_per_sm(const Plan& pl);

cudaError_t launch_map(const int2* xy, long long n_hits, long long* uq, long long* vq, int* status, cudaStream_t st);
cudaError_t launch_vote(const long long* uq, const long long* vq, const long long* off, long long n_events,
                        const hough_params& p, int16_t* acc, int* status, const TrigTable& trig, cudaStream_t st);
cudaError_t launch_peaks(const int16_t* acc, long long n_events, const hough_params& p, int* npeaks,
                         hough_peak* peaks, int* status, cudaStream_t st);
cudaError_t launch_select(const long long* uq, const long long* vq, const long long* off, long long n_events,
                          const hough_params& p, const int* npeaks, const hough_peak* peaks, uint8_t* mask,
                          int* nkept, int* status, const TrigTable& trig, cudaStream_t st);

cudaError_t launch_circles(const int* npeaks, const hough_peak* peaks, long long n_events, int n_theta, int n_rho,
                           int max_peaks, double b_tesla, float* circles, cudaStream_t st);
cudaError_t launch_rebase(long long* off, long long n, long long a0, cudaStream_t st);
cudaError_t launch_pack_peaks(const int* npeaks, const hough_peak* peaks, long long n_events, int max_peaks,
                              long long* peak_off, hough_peak* dense, cudaStream_t st);

cudaError_t launch_selftest_fpbin(const Plan& pl, const TrigTable& trig, unsigned long long seed, long long n,
                                  unsigned long long* out, cudaStream_t st);
cudaError_t launch_selftest_bin(int n_rho, long long lo, long long hi, unsigned long long* mismatch, cudaStream_t st);
cudaError_t launch_probe_atomics(int mode, int ctas_per_sm, int threads, int smem_bytes, int iters,
                                 unsigned long long* sink, cudaStream_t st);

// Records a CUDA error for hough_last_cuda_error (this host thread).
void note_cuda_error(cudaError_t e);

}  // namespace hgpu
