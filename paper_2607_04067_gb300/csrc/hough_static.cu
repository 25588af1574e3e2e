// hough_run_batched_static: the batched path for callers that cannot allocate device memory.
//
// Some callers of this library have no way to obtain a device workspace: a plain-C trigger
// process that links only libhough.so and whose input and output buffers were mapped once by
// the data-acquisition layer (for instance registered for direct transfer from the readout),
// or a real-time loop whose rules forbid any allocation after start-up because cudaMalloc may
// synchronise the device and make latency unbounded. They still hand in their inputs and
// outputs; this entry point takes the scratch the batched path needs (work-queue counter,
// event order, per-tile peak slots) from a fixed array compiled into the library instead of
// from a caller workspace.
//
// The array is a file-scope __device__ symbol, so every GPU that loads this library holds
// HOUGH_STATIC_SCRATCH_BYTES of it until the process exits. Host code cannot use the
// symbol's name as an address: the first call on each device looks the address up with
// cudaGetSymbolAddress (with that device current) and caches it. That first call should
// therefore happen before any stream capture. The cached address belongs to the device's
// primary context as it was at that first call: cudaDeviceReset destroys that context (and the
// array with it), so a process that resets a device must not call this entry point on that
// device afterwards. Every call shares the same array and leaves its
// contents behind, so calls that overlap on the GPU (other streams, other host threads) race
// and must be serialised by the caller. Everything that has to start at zero (the queue
// counter and the per-event tile tickets) is cleared by the validation kernel of each call.
#include <cstring>
#include <mutex>

#include "hough_internal.h"

namespace hgpu {

int make_plan(const hough_params* p, Plan& pl, int acc32);
void note_cuda_error(cudaError_t e);

namespace {

static __device__ __align__(256) unsigned char g_static_scratch[HOUGH_STATIC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of g_static_scratch on the current device (looked up once per device).
cudaError_t scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

int fail(cudaError_t e) {
  note_cuda_error(e);
  return HOUGH_ECUDA;
}

}  // namespace
}  // namespace hgpu

using namespace hgpu;

extern "C" int hough_run_batched_static(const int32_t* d_xy, int64_t n_hits, const int64_t* d_off, int64_t n_events,
                                        const hough_params* p, int32_t* d_npeaks, hough_peak* d_peaks,
                                        uint8_t* d_mask, int32_t* d_nkept, uint64_t* d_checksum, int32_t* d_status,
                                        void* stream) {
  if (!d_off || !d_status || n_hits < 0 || n_events < 0) return HOUGH_EINVAL;
  if (n_events > 0 && (!d_npeaks || !d_peaks || !d_nkept)) return HOUGH_EINVAL;
  if (n_hits > 0 && (!d_xy || !d_mask)) return HOUGH_EINVAL;
  if (((uintptr_t)d_xy & 7) || ((uintptr_t)d_peaks & 7)) return HOUGH_EINVAL;
  Plan pl;
  int rc = make_plan(p, pl, -1);
  if (rc) return rc;
  if ((long long)n_events * pl.tiles > 0x7fffffffLL) return HOUGH_EINVAL;
  const WsLayout wl = ws_layout(pl, n_events);
  if (wl.total > (size_t)HOUGH_STATIC_SCRATCH_BYTES) return HOUGH_EWORKSPACE;  // batch too large for the array
  void* base = nullptr;
  cudaError_t e = scratch_address(&base);
  if (e != cudaSuccess) return fail(e);
  char* ws = (char*)base;
  FusedIO io;
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
  bind_workspace(pl, wl, ws, io);
  io.n_items = n_events * (long long)pl.tiles;
  int* order = (int*)(ws + wl.order);
  cudaStream_t st = (cudaStream_t)stream;
  e = launch_prep(io.off, n_events, n_hits, d_status, io.queue, io.tickets, order, st);
  if (e != cudaSuccess) return fail(e);
  if (io.n_items == 0) return HOUGH_OK;
  int dev = 0, sms = 0;
  e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return fail(e);
  const int per_sm = fused_max_ctas_per_sm(pl);
  if (per_sm < 1) return HOUGH_ESMEM;
  long long grid = (long long)sms * per_sm;
  if (grid > io.n_items) grid = io.n_items;
  TrigTable trig;
  host_trig(p->n_theta, &trig);
  io.order = order;
  io.persistent = 1;
  e = launch_fused(pl, io, trig, (int)grid, st);
  return e == cudaSuccess ? HOUGH_OK : fail(e);
}
